// Stable bucketing (counting sort by key): offsets[b] = number of keys < b and order =
// the positions 0..n-1 grouped by key, ascending within each bucket - the inverted-file
// layout of section 2 ("groups the vectors into inverted lists"), lists in insertion
// order, and the member lists of k-means clusters.
//
// counts (atomics) -> exclusive scan (one block) -> scatter (atomic cursors, unordered)
// -> per-bucket ordering: buckets of up to SORT_CAP members are sorted in shared memory;
// larger ones are rebuilt by an order-preserving compaction over the key array.
#include <algorithm>

#include "common.cuh"
#include "ivf.cuh"

namespace gbk {

namespace {

constexpr int SORT_CAP = 8192;

__global__ void count_kernel(const int32_t* __restrict__ keys, int64_t n,
                             unsigned long long* __restrict__ counts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[keys[i]], 1ull);
}

// Exclusive scan of counts[0..nb) into offsets[0..nb] with a single 1024-thread block.
__global__ void __launch_bounds__(1024)
    scan_kernel(const unsigned long long* __restrict__ counts, int nb, int64_t* __restrict__ offsets,
                int64_t* __restrict__ cursor) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int b0 = t * per, b1 = min(nb, b0 + per);
  int64_t s = 0;
  for (int b = b0; b < b1; b++) s += (int64_t)counts[b];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = part[t] - s;  // exclusive prefix of this thread's range
  for (int b = b0; b < b1; b++) {
    offsets[b] = run;
    cursor[b] = run;
    run += (int64_t)counts[b];
  }
  if (t == 1023) offsets[nb] = part[1023];
}

__global__ void scatter_kernel(const int32_t* __restrict__ keys, int64_t n,
                               unsigned long long* __restrict__ cursor, int64_t* __restrict__ order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long pos = atomicAdd(&cursor[keys[i]], 1ull);
    order[pos] = i;
  }
}

// One block per bucket of at most SORT_CAP members: bitonic sort of its positions.
__global__ void __launch_bounds__(512)
    sort_small_kernel(const int64_t* __restrict__ offsets, int nb, int64_t* __restrict__ order,
                      int* __restrict__ big_count, int* __restrict__ big_list) {
  __shared__ uint32_t v[SORT_CAP];  // positions < 2^31
  const int b = blockIdx.x;
  const int64_t o0 = offsets[b], cnt = offsets[b + 1] - o0;
  if (cnt <= 1) return;
  if (cnt > SORT_CAP) {
    if (threadIdx.x == 0) big_list[atomicAdd(big_count, 1)] = b;
    return;
  }
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    v[i] = i < cnt ? (uint32_t)order[o0 + i] : 0xffffffffu;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const uint32_t a = v[lo], c = v[hi];
        if ((a > c) == asc) {
          v[lo] = c;
          v[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) order[o0 + i] = (int64_t)v[i];
}

// One block per large bucket: order-preserving compaction of {i : keys[i] == b}.
__global__ void __launch_bounds__(1024)
    compact_big_kernel(const int32_t* __restrict__ keys, int64_t n,
                       const int64_t* __restrict__ offsets, const int* __restrict__ big_count,
                       const int* __restrict__ big_list, int64_t* __restrict__ order) {
  __shared__ int warp_tot[32];
  __shared__ int64_t base_s;
  if ((int)blockIdx.x >= *big_count) return;
  const int b = big_list[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base_s = offsets[b];
  __syncthreads();
  for (int64_t i0 = 0; i0 < n; i0 += blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const bool hit = i < n && keys[i] == b;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      if (w < warp) before += warp_tot[w];
      total += warp_tot[w];
    }
    if (hit) order[base_s + before + __popc(bal & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (threadIdx.x == 0) base_s += total;
    __syncthreads();
  }
}

}  // namespace

gbk_status bucket_stable(const int32_t* keys, int64_t n, int nb, int64_t* offsets, int64_t* order,
                         cudaStream_t st) {
  ProfScope prof("bucket_stable", st);
  Scratch counts, cursor, big;
  gbk_status r;
  if ((r = counts.alloc(sizeof(unsigned long long) * (size_t)nb, st)) != GBK_OK) return r;
  if ((r = cursor.alloc(sizeof(int64_t) * (size_t)nb, st)) != GBK_OK) return r;
  if ((r = big.alloc(sizeof(int) * (size_t)(nb + 1), st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemsetAsync(counts.p, 0, sizeof(unsigned long long) * (size_t)nb, st));
  GBK_CUDA_CHECK(cudaMemsetAsync(big.p, 0, sizeof(int), st));
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256),
                                          (int64_t)device_info().sm_count * 16);
  if (n > 0) count_kernel<<<grid, 256, 0, st>>>(keys, n, counts.as<unsigned long long>());
  scan_kernel<<<1, 1024, 0, st>>>(counts.as<unsigned long long>(), nb, offsets,
                                  cursor.as<int64_t>());
  if (n > 0)
    scatter_kernel<<<grid, 256, 0, st>>>(keys, n, (unsigned long long*)cursor.p, order);
  int* bigc = big.as<int>();
  sort_small_kernel<<<nb, 512, 0, st>>>(offsets, nb, order, bigc, bigc + 1);
  // at most n / SORT_CAP buckets can exceed the capacity
  const int maxbig = (int)std::min<int64_t>(nb, n / SORT_CAP + 1);
  compact_big_kernel<<<maxbig, 1024, 0, st>>>(keys, n, offsets, bigc, bigc + 1, order);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace gbk
