// C ABI entry points: argument validation, error reporting and the scratch allocator.
// Every compute step runs in the library's kernels; there is no host fallback.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kselect.cuh"

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
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
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
  return kselect_run(vals, rows, len, k, largest != 0, D, I, as_stream(stream), nullptr);
}

gbk_status gbk_row_norms(const float* x, int64_t n, int32_t d, float* out, void* stream) {
  clear_error();
  GBK_REQUIRE(n >= 0 && d >= 1, "gbk_row_norms: bad sizes n=%lld d=%d", (long long)n, d);
  if (n == 0) return GBK_OK;
  GBK_REQUIRE(x && out, "gbk_row_norms: NULL pointer");
  return row_norms_run(x, n, d, out, as_stream(stream));
}

}  // extern "C"
