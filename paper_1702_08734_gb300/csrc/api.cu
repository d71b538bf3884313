// C ABI entry points: argument validation, error reporting and the scratch allocator.
// Every compute step runs in the library's kernels; there is no host fallback.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kselect.cuh"
#include "knn.cuh"
#include "ivf.cuh"

namespace gbk {

namespace {
thread_local char g_err[1024] = "";
std::mutex g_alloc_mu;
gbk_allocator g_alloc = {nullptr, nullptr, nullptr};
}  // namespace

gbk_status set_error(gbk_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

gbk_status clear_error() {
  g_err[0] = '\0';
  return GBK_OK;
}

// The library's own stream-ordered pool per device (the default pool is left as it is):
// it keeps up to 8 GiB of freed scratch mapped between calls instead of releasing it at
// every synchronisation, so a call that follows a synchronising one (host-buffer search,
// an end-to-end loop) does not map its scratch afresh.  0 on failure (then the default
// pool is used).
static cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  static bool failed[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev] && !failed[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      failed[dev] = true;
      return nullptr;
    }
    uint64_t keep = (uint64_t)8 << 30;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

void* scratch_alloc(size_t bytes, cudaStream_t stream, gbk_status* st) {
  gbk_allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  void* p = nullptr;
  if (a.alloc) {
    p = a.alloc(a.ctx, bytes, (void*)stream);
    if (!p) *st = set_error(GBK_ENOMEM, "installed allocator failed for %zu bytes", bytes);
    return p;
  }
  cudaMemPool_t pool = library_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, stream)
                       : cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    *st = set_error(GBK_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void scratch_free(void* p, cudaStream_t stream) {
  gbk_allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (a.alloc) {
    if (a.free) a.free(a.ctx, p, (void*)stream);
    return;
  }
  cudaFreeAsync(p, stream);
}

const DeviceInfo& device_info() {
  static thread_local DeviceInfo cache = {-1, 0, 0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (cache.device != dev) {
    cudaDeviceProp pr;
    cudaGetDeviceProperties(&pr, dev);
    cache.device = dev;
    cache.sm_count = pr.multiProcessorCount;
    cache.smem_optin = pr.sharedMemPerBlockOptin;
  }
  return cache;
}

gbk_status set_smem_limit(const void* kern, size_t bytes, bool max_carveout) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;  // (kernel, device) -> limit set
  int dev = 0;
  GBK_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({kern, dev});
  if (it != done.end() && it->second >= bytes) return GBK_OK;
  GBK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes));
  if (max_carveout)
    GBK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
  done[{kern, dev}] = bytes;
  return GBK_OK;
}

namespace {
struct ProfRec {
  char name[32];
  cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
thread_local const char* t_prof_suffix = "";
}  // namespace

ProfSuffix::ProfSuffix(const char* suffix) : prev(t_prof_suffix) { t_prof_suffix = suffix; }
ProfSuffix::~ProfSuffix() { t_prof_suffix = prev; }

ProfScope::ProfScope(const char* name, cudaStream_t st) : stream(st) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on || g_prof.size() >= 4096) return;
  ProfRec r;
  snprintf(r.name, sizeof(r.name), "%s%s", name, t_prof_suffix);
  if (cudaEventCreate(&r.e0) != cudaSuccess) return;
  if (cudaEventCreate(&r.e1) != cudaSuccess) return;
  cudaEventRecord(r.e0, st);
  g_prof.push_back(r);
  slot = (int)g_prof.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_prof.size()) cudaEventRecord(g_prof[slot].e1, stream);
}

uint32_t* device_status() {
  static std::mutex mu;
  static uint32_t* words[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!words[dev]) {
    uint32_t* p = nullptr;
    if (cudaMalloc(&p, sizeof(uint32_t)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(uint32_t)) != cudaSuccess) return nullptr;
    words[dev] = p;
  }
  return words[dev];
}

}  // namespace gbk

using namespace gbk;

extern "C" {

int32_t gbk_version(void) { return 100; }

const char* gbk_last_error(void) { return g_err; }

gbk_status gbk_set_allocator(const gbk_allocator* allocator) {
  clear_error();
  if (allocator && !allocator->alloc)
    return set_error(GBK_EINVAL, "gbk_set_allocator: alloc callback is NULL");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (allocator)
    g_alloc = *allocator;
  else
    g_alloc = gbk_allocator{nullptr, nullptr, nullptr};
  return GBK_OK;
}

gbk_status gbk_kselect(const float* vals, int64_t rows, int64_t len, int32_t k, int32_t largest,
                       float* D, int64_t* I, void* stream) {
  return gbk_kselect_ex(vals, rows, len, k, largest, D, I, nullptr, stream);
}

gbk_status gbk_kselect_ex(const float* vals, int64_t rows, int64_t len, int32_t k,
                          int32_t largest, float* D, int64_t* I, const gbk_kselect_opts* opts,
                          void* stream) {
  clear_error();
  GBK_REQUIRE(rows >= 0, "gbk_kselect: rows < 0");
  if (rows == 0) return GBK_OK;
  GBK_REQUIRE(len >= 1 && len < (int64_t(1) << 31), "gbk_kselect: len %lld out of [1, 2^31)",
              (long long)len);
  GBK_REQUIRE(k >= 1 && k <= GBK_MAX_K, "gbk_kselect: k=%d out of [1, %d]", k, GBK_MAX_K);
  GBK_REQUIRE(k <= len, "gbk_kselect: k=%d > len=%lld", k, (long long)len);
  GBK_REQUIRE(vals && D && I, "gbk_kselect: NULL pointer");
  GBK_REQUIRE(largest == 0 || largest == 1, "gbk_kselect: largest must be 0 or 1");
  GBK_REQUIRE(rows * (int64_t)k < (int64_t(1) << 40), "gbk_kselect: output too large");
  KselectTuning tu = kselect_default_tuning(rows, len, k);
  if (opts) {
    GBK_REQUIRE(opts->unroll == 0 || opts->unroll == 1 || opts->unroll == 4 || opts->unroll == 8,
                "gbk_kselect_ex: unroll must be 0, 1, 4 or 8");
    GBK_REQUIRE(opts->segments >= 0, "gbk_kselect_ex: segments < 0");
    if (opts->unroll) tu.unroll = opts->unroll;
    if (opts->segments) tu.segs = opts->segments;
  }
  return kselect_run(vals, rows, len, k, largest != 0, D, I, as_stream(stream), &tu);
}

void gbk_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
}

int32_t gbk_profile_read(char* names, float* ms, int32_t max_records) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int32_t n = 0;
  for (auto& r : g_prof) {
    cudaEventSynchronize(r.e1);
    if (n < max_records) {
      float t = 0.f;
      cudaEventElapsedTime(&t, r.e0, r.e1);
      if (ms) ms[n] = t;
      if (names) snprintf(names + 32 * n, 32, "%s", r.name);
    }
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
    n++;
  }
  g_prof.clear();
  return n < max_records ? n : max_records;
}

gbk_status gbk_device_status(void* stream) {
  clear_error();
  uint32_t* w = device_status();
  if (!w) return set_error(GBK_ECUDA, "device status word unavailable");
  GBK_CUDA_CHECK(cudaStreamSynchronize(as_stream(stream)));
  uint32_t v = 0;
  GBK_CUDA_CHECK(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
  if (v == 0) return GBK_OK;
  GBK_CUDA_CHECK(cudaMemset(w, 0, sizeof(uint32_t)));
  if (v & 1u) return set_error(GBK_ETIMEOUT, "a device-side wait gave up (status 0x%x)", v);
  return set_error(GBK_EDEVICE, "kernel status word 0x%x", v);
}

// Argument checks and options of gbk_knn_brute and gbk_knn_brute_host (`fn`: the
// entry point's name for the error messages).
static gbk_status knn_args(const char* fn, int64_t nq, int64_t nb, int32_t d, int32_t k,
                           int32_t metric, const void* xq, const void* xb, const void* D,
                           const void* I, const gbk_knn_opts* opts, KnnPlan* plan) {
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "%s: nq out of range", fn);
  GBK_REQUIRE(nb >= 1 && nb < (int64_t(1) << 31), "%s: nb out of range", fn);
  GBK_REQUIRE(d >= 1, "%s: d < 1", fn);
  GBK_REQUIRE(k >= 1 && k <= GBK_MAX_K && k <= nb, "%s: k=%d out of [1, min(nb, %d)]", fn, k,
              GBK_MAX_K);
  GBK_REQUIRE(metric == GBK_METRIC_L2 || metric == GBK_METRIC_IP, "%s: bad metric", fn);
  GBK_REQUIRE(nq == 0 || (xq && xb && D && I), "%s: NULL pointer", fn);
  if (opts) {
    GBK_REQUIRE(opts->precision >= GBK_PREC_FP32 && opts->precision <= GBK_PREC_TF32X3,
                "%s: bad precision", fn);
    GBK_REQUIRE(opts->chunks >= 0, "%s: chunks < 0", fn);
    GBK_REQUIRE(opts->prefilter >= -1 && opts->prefilter <= 1,
                "%s: prefilter must be -1, 0 or 1", fn);
    GBK_REQUIRE(opts->kprime == 0 || (opts->kprime >= k && opts->kprime <= GBK_MAX_K),
                "%s: kprime must be 0 or in [k, %d]", fn, GBK_MAX_K);
    plan->prec = opts->precision;
    plan->chunks = opts->chunks;
    plan->kprime = opts->kprime;
    plan->certified = opts->certified;
    plan->error_bound = opts->error_bound;
    plan->exact = opts->exact != 0;
    plan->prefilter = opts->prefilter;
  }
  return GBK_OK;
}

gbk_status gbk_knn_brute(const float* xq, int64_t nq, const float* xb, int64_t nb, int32_t d,
                         int32_t k, int32_t metric, float* D, int64_t* I,
                         const gbk_knn_opts* opts, void* stream) {
  clear_error();
  KnnPlan plan;
  gbk_status r = knn_args("gbk_knn_brute", nq, nb, d, k, metric, xq, xb, D, I, opts, &plan);
  if (r != GBK_OK || nq == 0) return r;
  return knn_run(xq, nq, xb, nb, d, k, metric, D, I, plan, as_stream(stream));
}

}  // extern "C"

struct gbk_knn_db {
  gbk::PreparedOperand B;  // the database operand in its precision
  const float* xb = nullptr;
  int64_t nb = 0;
  int d = 0, prec = 0;
};

extern "C" {

gbk_status gbk_knn_db_create(const float* xb, int64_t nb, int32_t d, int32_t precision,
                             gbk_knn_db** out, void* stream) {
  clear_error();
  GBK_REQUIRE(out, "gbk_knn_db_create: out is NULL");
  GBK_REQUIRE(xb, "gbk_knn_db_create: xb is NULL");
  GBK_REQUIRE(nb >= 1 && nb < (int64_t(1) << 31), "gbk_knn_db_create: nb out of range");
  GBK_REQUIRE(d >= 1, "gbk_knn_db_create: d < 1");
  GBK_REQUIRE(precision >= GBK_PREC_FP32 && precision <= GBK_PREC_TF32X3,
              "gbk_knn_db_create: bad precision");
  gbk_knn_db* db = new gbk_knn_db();
  db->xb = xb;
  db->nb = nb;
  db->d = d;
  db->prec = precision;
  const gbk_status r = prepare_database(xb, nb, d, precision, &db->B, as_stream(stream));
  if (r != GBK_OK) {
    delete db;
    return r;
  }
  *out = db;
  return GBK_OK;
}

gbk_status gbk_knn_db_search(const gbk_knn_db* db, const float* xq, int64_t nq, int32_t k,
                             int32_t metric, float* D, int64_t* I, const gbk_knn_opts* opts,
                             void* stream) {
  clear_error();
  GBK_REQUIRE(db, "gbk_knn_db_search: db is NULL");
  KnnPlan plan;
  plan.prec = db->prec;
  gbk_status r = knn_args("gbk_knn_db_search", nq, db->nb, db->d, k, metric, xq, db->xb, D, I,
                          opts, &plan);
  if (r != GBK_OK || nq == 0) return r;
  GBK_REQUIRE(!opts || opts->precision == db->prec,
              "gbk_knn_db_search: options ask for precision %d, the database is prepared in %d",
              opts ? opts->precision : 0, db->prec);
  return knn_run_prepared(xq, nq, db->xb, db->B, db->nb, db->d, k, metric, D, I, plan,
                          as_stream(stream));
}

void gbk_knn_db_destroy(gbk_knn_db* db, void* stream) {
  if (!db) return;
  cudaStream_t st = as_stream(stream);
  db->B.data.stream = st;  // freed stream-ordered on the caller's stream
  db->B.norms.stream = st;
  db->B.scale.stream = st;
  delete db;
}

gbk_status gbk_knn_brute_host(const float* xq, int64_t nq, const float* xb, int64_t nb,
                              int32_t d, int32_t k, int32_t metric, float* D, int64_t* I,
                              const gbk_knn_opts* opts, void* stream) {
  clear_error();
  KnnPlan plan;
  gbk_status r =
      knn_args("gbk_knn_brute_host", nq, nb, d, k, metric, xq, xb, D, I, opts, &plan);
  if (r != GBK_OK || nq == 0) return r;
  GBK_REQUIRE(!plan.certified && !plan.error_bound,
              "gbk_knn_brute_host: certified / error_bound outputs are device arrays; use "
              "gbk_knn_brute");
  return knn_host_run(xq, nq, xb, nb, d, k, metric, D, I, plan, as_stream(stream));
}

gbk_status gbk_merge_topk(const float* D_parts, const int64_t* I_parts, int32_t nparts,
                          int64_t nq, int32_t k_in, int32_t k, int32_t largest, float* D,
                          int64_t* I, void* stream) {
  clear_error();
  GBK_REQUIRE(nparts >= 1 && k_in >= 1 && k >= 1 && k <= GBK_MAX_K,
              "gbk_merge_topk: bad sizes");
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "gbk_merge_topk: nq out of range");
  GBK_REQUIRE((int64_t)nparts * k_in < (int64_t(1) << 31), "gbk_merge_topk: too many entries");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(D_parts && I_parts && D && I, "gbk_merge_topk: NULL pointer");
  return merge_parts_run(D_parts, I_parts, nparts, nq, k_in, k, largest != 0, D, I,
                         as_stream(stream));
}

gbk_status gbk_pairwise_distances(const float* xq, int64_t nq, const float* xb, int64_t nb,
                                  int32_t d, int32_t metric, int32_t precision, float* out,
                                  int64_t ldo, void* stream) {
  clear_error();
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "gbk_pairwise_distances: nq out of range");
  GBK_REQUIRE(nb >= 1 && nb < (int64_t(1) << 31), "gbk_pairwise_distances: nb out of range");
  GBK_REQUIRE(d >= 1 && ldo >= nb, "gbk_pairwise_distances: bad d or ldo");
  GBK_REQUIRE(metric == GBK_METRIC_L2 || metric == GBK_METRIC_IP,
              "gbk_pairwise_distances: bad metric");
  GBK_REQUIRE(precision >= GBK_PREC_FP32 && precision <= GBK_PREC_TF32X3,
              "gbk_pairwise_distances: bad precision");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(xq && xb && out, "gbk_pairwise_distances: NULL pointer");
  cudaStream_t st = as_stream(stream);
  PreparedOperand Q, B;
  gbk_status r;
  const int64_t ntiles = (nb + 127) / 128;
  if ((r = prepare_operand(xq, nq, d, precision, nq, 0.f, &Q, st)) != GBK_OK) return r;
  if ((r = prepare_operand(xb, nb, d, precision, ntiles * 128, 0.f, &B, st)) != GBK_OK) return r;
  return pairwise_run(Q, B, metric == GBK_METRIC_IP, out, ldo, st);
}

gbk_status gbk_kmeans(const float* x, int64_t n, int32_t d, int32_t nc, int32_t niter,
                      const int64_t* init_idx, float* centroids, double* objective,
                      int64_t* n_split, int32_t direct_assign, void* stream) {
  clear_error();
  GBK_REQUIRE(x && init_idx && centroids, "gbk_kmeans: NULL argument");
  GBK_REQUIRE(n >= 1 && n < (int64_t(1) << 31) && d >= 1 && nc >= 1 && nc <= n && niter >= 0,
              "gbk_kmeans: bad sizes");
  for (int i = 0; i < nc; i++)
    GBK_REQUIRE(init_idx[i] >= 0 && init_idx[i] < n, "gbk_kmeans: init_idx out of range");
  cudaStream_t st = as_stream(stream);
  Scratch ii;
  gbk_status r;
  if ((r = ii.alloc(sizeof(int64_t) * (size_t)nc, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(ii.p, init_idx, sizeof(int64_t) * (size_t)nc,
                                 cudaMemcpyHostToDevice, st));
  r = kmeans_run(x, n, d, d, nc, niter, ii.as<int64_t>(), centroids, objective,
                 reinterpret_cast<long long*>(n_split), direct_assign != 0, st);
  if (r == GBK_OK) GBK_CUDA_CHECK(cudaStreamSynchronize(st));  // host init array reused
  return r;
}

gbk_status gbk_kselect_static(const float* vals, int64_t rows, int64_t len, int32_t k,
                              int32_t largest, int32_t segments, float* D, int64_t* I,
                              void* stream) {
  clear_error();
  GBK_REQUIRE(rows >= 0, "gbk_kselect_static: rows < 0");
  if (rows == 0) return GBK_OK;
  GBK_REQUIRE(len >= 1 && len < (int64_t(1) << 31), "gbk_kselect_static: len out of [1, 2^31)");
  GBK_REQUIRE(k >= 1 && k <= GBK_MAX_K && k <= len, "gbk_kselect_static: k=%d out of [1, min(len, %d)]",
              k, GBK_MAX_K);
  GBK_REQUIRE(vals && D && I, "gbk_kselect_static: NULL pointer");
  GBK_REQUIRE(largest == 0 || largest == 1, "gbk_kselect_static: largest must be 0 or 1");
  GBK_REQUIRE(segments >= 0, "gbk_kselect_static: segments < 0");
  return kselect_static_run(vals, rows, len, k, largest != 0, segments, D, I, as_stream(stream));
}

gbk_status gbk_row_norms(const float* x, int64_t n, int32_t d, float* out, void* stream) {
  clear_error();
  GBK_REQUIRE(n >= 0 && d >= 1, "gbk_row_norms: bad sizes n=%lld d=%d", (long long)n, d);
  if (n == 0) return GBK_OK;
  GBK_REQUIRE(x && out, "gbk_row_norms: NULL pointer");
  return row_norms_run(x, n, d, out, as_stream(stream));
}

}  // extern "C"
