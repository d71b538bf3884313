// Self-test of the failure-detection path: a bounded device-side wait that nothing will
// satisfy gives up after its limit, records the timeout in the device status word and
// returns, so that the context stays usable and the host learns of it through
// gbk_device_status.  The same bounded wait (sm100.cuh) guards every mbarrier wait of the
// library's kernels.
#include "common.cuh"
#include "sm100.cuh"

namespace gbk {
namespace {

// One thread: an mbarrier expecting one arrival that never comes, waited on for at most
// limit_ns of %globaltimer time.
__global__ void bounded_wait_kernel(uint64_t limit_ns, uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  sm100::mbar_init(&bar, 1);
  sm100::fence_mbar_init();
  const uint64_t t0 = sm100::globaltimer();
  for (;;) {
    if (sm100::mbar_try_wait(&bar, 0)) return;  // not reached: nothing arrives
    if (sm100::globaltimer() - t0 > limit_ns) {
      atomicOr(status, sm100::STATUS_TIMEOUT);
      return;
    }
  }
}

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" {

gbk_status gbk_selftest_wait_timeout(int64_t limit_ns, void* stream) {
  clear_error();
  GBK_REQUIRE(limit_ns >= 1000 && limit_ns <= (int64_t)sm100::WAIT_LIMIT_NS,
              "gbk_selftest_wait_timeout: limit out of [1 us, 2 s]");
  uint32_t* status = device_status();
  if (!status) return set_error(GBK_ECUDA, "device status word unavailable");
  bounded_wait_kernel<<<1, 32, 0, as_stream(stream)>>>((uint64_t)limit_ns, status);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // extern "C"
