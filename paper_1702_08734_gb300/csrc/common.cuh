// Shared host-side plumbing of the CUDA library: status codes, the thread-local error
// message, the scratch allocator hook and cached device properties.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
#include <string>

#include "../../include/gbknn.h"

namespace gbk {

// Records a message for gbk_last_error() and returns the status.
gbk_status set_error(gbk_status st, const char* fmt, ...);
gbk_status clear_error();

// Scratch memory from the installed allocator (default: the stream-ordered pool).
void* scratch_alloc(size_t bytes, cudaStream_t stream, gbk_status* st);
void scratch_free(void* p, cudaStream_t stream);

struct DeviceInfo {
  int device;
  int sm_count;
  size_t smem_optin;
};
const DeviceInfo& device_info();

// Per-device error word that kernels set instead of trapping (bit 0: a bounded wait
// gave up).  Allocated and zeroed on first use for the current device.
uint32_t* device_status();

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device (and, with
// max_carveout, prefer the largest shared-memory carveout).  Done once per (kernel, device)
// and per larger request; safe to call from several host threads.
gbk_status set_smem_limit(const void* kern, size_t bytes, bool max_carveout = false);
template <class F>
inline gbk_status set_smem_limit(F* kern, size_t bytes, bool max_carveout = false) {
  return set_smem_limit(reinterpret_cast<const void*>(kern), bytes, max_carveout);
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Optional per-kernel timing (gbk_profile_*): when enabled, a scope records a CUDA event
// pair on the launch stream around the kernel(s) it covers.
struct ProfScope {
  int slot = -1;
  cudaStream_t stream = nullptr;
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
};
// While one is alive on a host thread, the names its ProfScopes record carry `suffix`
// (e.g. the kernels of a helper pass told apart from the main pass's).
struct ProfSuffix {
  const char* prev;
  explicit ProfSuffix(const char* suffix);
  ~ProfSuffix();
};

// RAII scratch buffer (freed stream-ordered at scope exit).
struct Scratch {
  void* p = nullptr;
  cudaStream_t stream = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  gbk_status alloc(size_t bytes, cudaStream_t s) {
    gbk_status st = GBK_OK;
    stream = s;
    p = bytes ? scratch_alloc(bytes, s, &st) : nullptr;
    return st;
  }
  ~Scratch() {
    if (p) scratch_free(p, stream);
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

}  // namespace gbk

#define GBK_CUDA_CHECK(expr)                                                                 \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return ::gbk::set_error(GBK_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #expr,          \
                              cudaGetErrorString(e_));                                       \
  } while (0)

#define GBK_LAUNCH_CHECK()                                                                   \
  do {                                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess)                                                                   \
      return ::gbk::set_error(GBK_ECUDA, "%s:%d launch: %s", __FILE__, __LINE__,            \
                              cudaGetErrorString(e_));                                       \
  } while (0)

#define GBK_TRY(expr)                                                                        \
  do {                                                                                       \
    const gbk_status s_ = (expr);                                                            \
    if (s_ != GBK_OK) return s_;                                                             \
  } while (0)

#define GBK_REQUIRE(cond, ...)                                                               \
  do {                                                                                       \
    if (!(cond)) return ::gbk::set_error(GBK_EINVAL, __VA_ARGS__);                           \
  } while (0)
