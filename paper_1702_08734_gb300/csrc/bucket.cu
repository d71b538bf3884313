// Stable bucketing (counting sort by key): offsets[b] = number of keys < b and order =
// the positions 0..n-1 grouped by key, ascending within each bucket - the inverted-file
// layout of section 2 ("groups the vectors into inverted lists"), lists in insertion
// order, and the member lists of k-means clusters.
//
// Many buckets: counts (atomics) -> exclusive scan (one block) -> scatter (atomic cursors,
// unordered) -> per-bucket ordering: buckets of up to SORT_CAP members are sorted in shared
// memory; larger ones are rebuilt by an order-preserving compaction over the key array.
// Few buckets (<= 4,096): per-tile histograms, a bucket-major scan of them, and a stable
// scatter from each tile sorted by (key, position) in shared memory.
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

// ---- tiled path (few buckets): per-tile histograms, a bucket-major scan, and a stable
// scatter from a sorted tile.  No global atomics, so few large buckets cost no contention.
constexpr int TILE = 2048, TILE_T = 256, TILE_BITS = 11;

__global__ void __launch_bounds__(TILE_T)
    tile_hist_kernel(const int32_t* __restrict__ keys, int64_t n, int nb, int ntiles,
                     uint32_t* __restrict__ H) {
  extern __shared__ uint32_t h[];  // [nb]
  const int tile = blockIdx.x;
  for (int b = threadIdx.x; b < nb; b += TILE_T) h[b] = 0u;
  __syncthreads();
  const int64_t i0 = (int64_t)tile * TILE;
  for (int j = threadIdx.x; j < TILE; j += TILE_T)
    if (i0 + j < n) atomicAdd(&h[keys[i0 + j]], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += TILE_T) H[(int64_t)b * ntiles + tile] = h[b];
}

// Block-wide exclusive scan of one value per thread (TILE_T threads); returns the total.
__device__ __forceinline__ int64_t block_exscan(int64_t v, int64_t* sh, int64_t& excl) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < TILE_T; o <<= 1) {
    const int64_t u = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += u;
    __syncthreads();
  }
  excl = sh[t] - v;
  const int64_t tot = sh[TILE_T - 1];
  __syncthreads();
  return tot;
}

// One block per bucket: the bucket's total over all tiles.
__global__ void __launch_bounds__(TILE_T)
    row_total_kernel(const uint32_t* __restrict__ H, int ntiles,
                     unsigned long long* __restrict__ tot) {
  __shared__ int64_t sh[TILE_T];
  const int b = blockIdx.x;
  int64_t s = 0;
  for (int t = threadIdx.x; t < ntiles; t += TILE_T) s += H[(int64_t)b * ntiles + t];
  int64_t excl;
  const int64_t all = block_exscan(s, sh, excl);
  if (threadIdx.x == 0) tot[b] = (unsigned long long)all;
}

// One block per bucket: H[b][t] <- offsets[b] + sum of H[b][t'] for t' < t (global base of
// bucket b's members in tile t).  Rows are scanned in per-thread runs of consecutive tiles.
__global__ void __launch_bounds__(TILE_T)
    row_scan_kernel(uint32_t* __restrict__ H, int ntiles, const int64_t* __restrict__ offsets,
                    int64_t* __restrict__ base) {
  __shared__ int64_t sh[TILE_T];
  const int b = blockIdx.x;
  const int per = (ntiles + TILE_T - 1) / TILE_T;
  const int t0 = threadIdx.x * per, t1 = min(ntiles, t0 + per);
  int64_t s = 0;
  for (int t = t0; t < t1; t++) s += H[(int64_t)b * ntiles + t];
  int64_t run;
  block_exscan(s, sh, run);
  run += offsets[b];
  for (int t = t0; t < t1; t++) {
    const int64_t c = H[(int64_t)b * ntiles + t];
    base[(int64_t)b * ntiles + t] = run;
    run += c;
  }
}

// Per tile: sort (key << 11 | position in tile) in shared memory; an element's rank among
// the tile's members of its bucket is its distance to the start of its key's run.
__global__ void __launch_bounds__(TILE_T)
    tile_scatter_kernel(const int32_t* __restrict__ keys, int64_t n, int nb, int ntiles,
                        const int64_t* __restrict__ base, int64_t* __restrict__ order) {
  __shared__ uint32_t v[TILE];
  extern __shared__ uint32_t start[];  // [nb] first sorted index of each key in the tile
  const int tile = blockIdx.x;
  const int64_t i0 = (int64_t)tile * TILE;
  for (int j = threadIdx.x; j < TILE; j += TILE_T)
    v[j] = i0 + j < n ? ((uint32_t)keys[i0 + j] << TILE_BITS) | (uint32_t)j : 0xffffffffu;
  __syncthreads();
  for (int size = 2; size <= TILE; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < TILE / 2; t += TILE_T) {
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
  for (int j = threadIdx.x; j < TILE; j += TILE_T) {
    const uint32_t e = v[j];
    if (e != 0xffffffffu && (j == 0 || (v[j - 1] >> TILE_BITS) != (e >> TILE_BITS)))
      start[e >> TILE_BITS] = (uint32_t)j;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < TILE; j += TILE_T) {
    const uint32_t e = v[j];
    if (e == 0xffffffffu) continue;
    const uint32_t key = e >> TILE_BITS;
    order[base[(int64_t)key * ntiles + tile] + (j - (int)start[key])] =
        i0 + (int64_t)(e & (TILE - 1));
  }
}

}  // namespace

static gbk_status bucket_tiled(const int32_t* keys, int64_t n, int nb, int64_t* offsets,
                               int64_t* order, cudaStream_t st) {
  const int ntiles = (int)((n + TILE - 1) / TILE);
  Scratch H, base, tot, cursor;
  gbk_status r;
  if ((r = H.alloc(sizeof(uint32_t) * (size_t)nb * ntiles, st)) != GBK_OK) return r;
  if ((r = base.alloc(sizeof(int64_t) * (size_t)nb * ntiles, st)) != GBK_OK) return r;
  if ((r = tot.alloc(sizeof(unsigned long long) * (size_t)nb, st)) != GBK_OK) return r;
  if ((r = cursor.alloc(sizeof(int64_t) * (size_t)nb, st)) != GBK_OK) return r;
  const size_t hs = sizeof(uint32_t) * (size_t)nb;
  tile_hist_kernel<<<ntiles, TILE_T, hs, st>>>(keys, n, nb, ntiles, H.as<uint32_t>());
  row_total_kernel<<<nb, TILE_T, 0, st>>>(H.as<uint32_t>(), ntiles, tot.as<unsigned long long>());
  scan_kernel<<<1, 1024, 0, st>>>(tot.as<unsigned long long>(), nb, offsets, cursor.as<int64_t>());
  row_scan_kernel<<<nb, TILE_T, 0, st>>>(H.as<uint32_t>(), ntiles, offsets, base.as<int64_t>());
  tile_scatter_kernel<<<ntiles, TILE_T, hs, st>>>(keys, n, nb, ntiles, base.as<int64_t>(), order);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status bucket_stable(const int32_t* keys, int64_t n, int nb, int64_t* offsets, int64_t* order,
                         cudaStream_t st) {
  ProfScope prof("bucket_stable", st);
  // few buckets (k-means with up to 4,096 clusters, work-order keys): the tiled path
  if (n > 0 && nb <= 4096 && (int64_t)nb * ((n + TILE - 1) / TILE) <= (int64_t(1) << 24))
    return bucket_tiled(keys, n, nb, offsets, order, st);
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
