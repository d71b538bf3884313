// Squared row norms ||x_i||^2: the two precomputable terms of Eq. (2) (section 2,
// "Exact search").  One warp per row, 16-byte loads when the row allows them, a
// fixed-order float32 sum (lane partials, then a butterfly).
#include "common.cuh"
#include "kselect.cuh"

namespace gbk {

namespace {

__global__ void row_norms_kernel(const float* __restrict__ x, int64_t n, int d,
                                 float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* p = x + row * d;
  float s = 0.f;
  if ((d & 3) == 0 && (((uintptr_t)p) & 15) == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    for (int i = lane; i < d / 4; i += 32) {
      float4 v = __ldg(p4 + i);
      s = fmaf(v.x, v.x, s);
      s = fmaf(v.y, v.y, s);
      s = fmaf(v.z, v.z, s);
      s = fmaf(v.w, v.w, s);
    }
  } else {
    for (int i = lane; i < d; i += 32) s = fmaf(p[i], p[i], s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = s;
}

}  // namespace

gbk_status row_norms_run(const float* x, int64_t n, int d, float* out, cudaStream_t stream) {
  if (n == 0) return GBK_OK;
  const int warps = 8;
  const int64_t blocks = (n + warps - 1) / warps;
  row_norms_kernel<<<(unsigned)blocks, warps * 32, 0, stream>>>(x, n, d, out);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace gbk
